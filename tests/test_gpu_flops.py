"""The engine's per-launch FLOP bookkeeping (what the benchmark divides by
device time) against the oracle's independent count of the algorithmic
FLOPs of the transfer-matrix overlap (Section 2.1).  Both are sums of
integers below 2^53, so they must agree exactly."""
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


@pytest.fixture(scope="module", params=["fp64", "tf32x3"])
def ctx(td, request):
    c = td.Context(request.param)
    c.stats_enable(True)
    yield c
    c.close()


def _engine_flops(td, ctx, bra_o, ket_o):
    bra = td.mps_import(ctx, bra_o.tensors, bra_o.labels)
    ket = td.mps_import(ctx, ket_o.tensors, ket_o.labels)
    ctx.stats_reset()
    got = td.overlap(ctx, bra, ket)
    st = ctx.stats()
    assert st["wstage"]["flops"] == 0
    ref = om.overlap(bra_o, ket_o)
    assert abs(got - ref) < 1e-10 * max(1.0, abs(ref))
    return st["gemm"]["flops"] + st["gemm_fp64"]["flops"]


@pytest.mark.parametrize("L,N,Dk,Db", [(16, 15, 256, 256), (16, 15, 256, 96), (8, 7, 40, 25)])
def test_overlap_flops_random_mps(td, ctx, L, N, Dk, Db):
    A, q = synth.random_mps(L, N, 1, Dk, seed=1)
    B, qb = synth.random_mps(L, N, 1, Db, seed=2)
    ket, bra = om.from_arrays(A, q), om.from_arrays(B, qb)
    assert _engine_flops(td, ctx, bra, ket) == om.overlap_flops(bra, ket)
    assert _engine_flops(td, ctx, ket, bra) == om.overlap_flops(ket, bra)


def test_overlap_flops_sparse_superpositions(td, ctx):
    rng = np.random.default_rng(5)
    dets = fci.basis(5, 3, 2)
    for _ in range(6):
        states = []
        for _side in range(2):
            pick = rng.choice(len(dets), size=3, replace=False)
            vec = np.zeros(len(dets), dtype=np.complex128)
            vec[pick] = rng.normal(size=3) + 1j * rng.normal(size=3)
            states.append(om.from_fock(om.sector_to_fock(vec, dets, 5), 5))
        bra, ket = states
        assert _engine_flops(td, ctx, bra, ket) == om.overlap_flops(bra, ket)


def test_overlap_flops_determinants(td, ctx):
    rng = np.random.default_rng(9)
    for _ in range(4):
        da = [int(x) for x in rng.permutation([3, 3, 1, 2, 0, 0, 0, 0])]
        db = [int(x) for x in rng.permutation([3, 3, 1, 2, 0, 0, 0, 0])]
        bra, ket = om.from_determinant(db), om.from_determinant(da)
        assert _engine_flops(td, ctx, bra, ket) == om.overlap_flops(bra, ket)
