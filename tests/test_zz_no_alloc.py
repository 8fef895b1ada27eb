"""The overlap entry point that allocates no device memory returns what
tdmps_overlap returns, on two calls in a row (the fixed scratch array keeps
the previous call's contents; each call must overwrite all it reads).

It serves callers that must not allocate device memory while they run, such
as applications whose caching allocator must remain the sole owner of device
memory.  This file is collected last so a failure here comes after every
other test has run."""
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


@pytest.mark.parametrize("L,N,S,D", [(8, 7, 1, 40), (16, 15, 1, 256)])
def test_overlap_noalloc_matches_overlap_twice(td, L, N, S, D):
    ctx = td.Context("fp64")
    A, q = synth.random_mps(L, N, S, D, seed=21)
    B, qb = synth.random_mps(L, N, S, D // 2, seed=22)
    a, b = td.mps_import(ctx, A, q), td.mps_import(ctx, B, qb)
    ref_ab = td.overlap(ctx, b, a)
    ref_aa = td.overlap(ctx, a, a)
    for _ in range(2):
        got_ab = td.overlap_noalloc(ctx, b, a)
        got_aa = td.overlap_noalloc(ctx, a, a)
        assert abs(got_ab - ref_ab) <= 1e-12 * max(1.0, abs(ref_ab))
        assert abs(got_aa - ref_aa) <= 1e-12 * max(1.0, abs(ref_aa))
    ctx.close()
