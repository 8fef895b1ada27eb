"""GPU: the instance batch (many independent evolutions of uneven size on
worker streams) gives the results of separate integrator calls, the oracle's
for one item, and isolates a failing item."""
import numpy as np
import pytest

import synth
from oracle import fci
from oracle import mps as om

pytestmark = pytest.mark.gpu

ITEMS = [(4, 4, 0, 16, 31), (5, 5, 1, 24, 32), (6, 6, 0, 32, 33), (5, 4, 0, 20, 34),
         (6, 5, -1, 28, 35), (4, 3, 1, 12, 36)]


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
    c.set_schedule(1, 1)
    yield c
    c.close()


def _vec(m):
    t, q = m.export()
    return om.to_fock(om.from_arrays(t, q))


def _setup(td, ctx):
    mpos, a, b, raw = [], [], [], []
    for L, n, sz, D, seed in ITEMS:
        I = synth.make_integrals(L, seed=seed)
        A, q = synth.random_mps(L, n, sz, D, seed=seed)
        mpos.append(td.build_mpo(ctx, I.h, I.eri, n_elec=n))
        a.append(td.mps_import(ctx, A, q))
        b.append(td.mps_import(ctx, A, q))
        raw.append((I, A, q))
    return mpos, a, b, raw


@pytest.mark.parametrize("method", ["rk4", "krylov"])
def test_batch_equals_separate_calls(td, ctx, method):
    mpos, a, b, raw = _setup(td, ctx)
    Ds = [it[3] for it in ITEMS]
    dt, steps = 0.01, 2 if method == "rk4" else 1
    st = td.evolve_batch(ctx, mpos, a, dt, steps, Ds, method=method, m=4, n_workers=3)
    assert (st == 0).all()
    for k in range(len(ITEMS)):
        for _ in range(steps):
            if method == "rk4":
                td.rk4_step(ctx, mpos[k], b[k], dt, Ds[k])
            else:
                td.krylov_step(ctx, mpos[k], b[k], dt, 4, True, Ds[k])
        va, vb = _vec(a[k]), _vec(b[k])
        assert np.linalg.norm(va - vb) <= 1e-11 * np.linalg.norm(vb)


def test_batch_item_matches_oracle(td, ctx):
    mpos, a, _, raw = _setup(td, ctx)
    td.evolve_batch(ctx, mpos, a, 0.01, 2, [it[3] for it in ITEMS], method="rk4", n_workers=4)
    k = 4
    L, n, sz, D, _ = ITEMS[k]
    I, A, q = raw[k]
    sys_ = om.System.build(I.h, I.eri, (n + sz) // 2, (n - sz) // 2)
    sch = om.Schedule(D=D, eps=0.0, n_two_site=1, n_one_site=1)
    ref = om.from_arrays(A, q)
    for _ in range(2):
        ref = om.rk4_step(sys_, ref, 0.01, sch)
    vr = sys_.vec(ref)
    vg = _vec(a[k])[sys_.fidx]
    fid = abs(np.vdot(vr, vg)) / (np.linalg.norm(vr) * np.linalg.norm(vg))
    assert 1 - fid < 1e-12
    assert abs(np.linalg.norm(vg) - np.linalg.norm(vr)) < 1e-10


def test_failing_item_is_isolated(td, ctx):
    mpos, a, _, raw = _setup(td, ctx)
    # a full orbital set (every orbital doubly occupied) has a one-dimensional
    # sector: the Krylov overlap matrix of m = 3 vectors has rank 1
    I2 = synth.make_integrals(2, seed=40)
    full = td.mps_from_determinant(ctx, [3, 3])
    mfull = td.build_mpo(ctx, I2.h, I2.eri, n_elec=4)
    states = a[:2] + [full] + a[2:4]
    mp = mpos[:2] + [mfull] + mpos[2:4]
    Ds = [16, 24, 4, 32, 20]
    before = _vec(full)
    st = td.evolve_batch(ctx, mp, states, 0.02, 1, Ds, method="krylov", m=3, n_workers=2,
                         raise_on_error=False)
    assert st[2] != 0 and (np.delete(st, 2) == 0).all()
    assert np.allclose(_vec(full), before)
    with pytest.raises(td.TdmpsError) as e:
        td.evolve_batch(ctx, mp, states, 0.02, 1, Ds, method="krylov", m=3, n_workers=2)
    assert "batch item 2" in str(e.value)
