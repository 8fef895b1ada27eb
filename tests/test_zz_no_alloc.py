"""The overlap entry point that allocates no device memory returns what
tdmps_overlap returns, on two calls in a row (the fixed scratch array keeps
the previous call's contents; each call must overwrite all it reads).

It serves callers that must not allocate device memory while they run, such
as applications whose caching allocator must remain the sole owner of device
memory.  The tests also watch the device's default memory pool (where the
library's stream-ordered allocations come from) while it runs, and check that
a pair too large for the fixed scratch is refused before any work starts and
leaves the context usable.  This file is collected last so a failure here
comes after every other test has run."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

# CUmemPool_attribute values of the CUDA driver API
USED_MEM_CURRENT, USED_MEM_HIGH = 7, 8


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


class _Pool:
    """The default memory pool of device 0 through the driver API."""

    def __init__(self):
        self.cu = ctypes.CDLL("libcuda.so.1")
        self.pool = ctypes.c_void_p()
        dev = ctypes.c_int()
        assert self.cu.cuDeviceGet(ctypes.byref(dev), 0) == 0
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def get(self, attr):
        v = ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):
        zero = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, USED_MEM_HIGH, ctypes.byref(zero)) == 0


def test_overlap_noalloc_leaves_the_device_pool_unchanged(td):
    import torch
    ctx = td.Context("fp64")
    A, q = synth.random_mps(16, 15, 1, 256, seed=23)
    B, qb = synth.random_mps(16, 15, 1, 200, seed=24)
    a, b = td.mps_import(ctx, A, q), td.mps_import(ctx, B, qb)
    ref = td.overlap(ctx, b, a)          # allocates (and frees) its environments
    torch.cuda.synchronize()
    pool = _Pool()
    pool.reset_high()
    before = pool.get(USED_MEM_CURRENT)
    for _ in range(2):
        got = td.overlap_noalloc(ctx, b, a)
        assert abs(got - ref) <= 1e-12 * max(1.0, abs(ref))
    torch.cuda.synchronize()
    assert pool.get(USED_MEM_HIGH) <= before
    # the regular entry point does allocate from that pool (the watch works)
    pool.reset_high()
    td.overlap(ctx, b, a)
    torch.cuda.synchronize()
    assert pool.get(USED_MEM_HIGH) > before
    ctx.close()


def _wide_pair():
    """L = 4, N = 4, 2S_z = 0 with deliberately redundant bonds of 600 / 1100
    vectors per sector: the intermediate E A at site 1 has 2 x 600 x 1100
    complex entries, more than the 1 M of the fixed scratch (16 MB)."""
    dims = [{(0, 0): 1}, {(1, 1): 600, (1, -1): 600}, {(2, 0): 1100},
            {(3, 1): 600, (3, -1): 600}, {(4, 0): 1}]
    qs = [(0, 0), (1, 1), (1, -1), (2, 0)]
    rng = np.random.default_rng(5)
    labels = [np.array([q for q, d in b.items() for _ in range(d)], dtype=np.int64).reshape(-1, 2)
              for b in dims]
    tensors = []
    for i in range(4):
        ql, qr = labels[i], labels[i + 1]
        A = np.zeros((len(ql), 4, len(qr)), dtype=np.complex128)
        for s, c in enumerate(qs):
            for a in range(len(ql)):
                tgt = ql[a] + np.array(c)
                cols = np.where(np.all(qr == tgt, axis=1))[0]
                if len(cols):
                    A[a, s, cols] = (rng.standard_normal(len(cols)) +
                                     1j * rng.standard_normal(len(cols))) / np.sqrt(len(cols))
        tensors.append(A)
    return tensors, labels


def test_overlap_noalloc_refuses_a_pair_beyond_the_scratch(td):
    ctx = td.Context("fp64")
    T, q = _wide_pair()
    w = td.mps_import(ctx, T, q)
    with pytest.raises(td.TdmpsError) as e:
        td.overlap_noalloc(ctx, w, w)
    assert e.value.name == "INVALID_ARG"
    # refused before any work: the context still computes both overlaps
    A, qa = synth.random_mps(8, 7, 1, 40, seed=25)
    a = td.mps_import(ctx, A, qa)
    ref = td.overlap(ctx, a, a)
    assert abs(td.overlap_noalloc(ctx, a, a) - ref) <= 1e-12 * abs(ref)
    ctx.close()
