"""The seeded input generators (shared by the oracle and the GPU tests):
random MPS structure and integral symmetries (no method arithmetic here)."""
import numpy as np
import pytest

import synth

SITE_Q = np.array(synth.states.SITE_CHARGE)


@pytest.mark.parametrize("L,N,S,D,seed", [(6, 5, 1, 12, 0), (8, 8, 0, 40, 3), (16, 15, 1, 256, 1)])
def test_random_mps_structure(L, N, S, D, seed):
    A, q = synth.random_mps(L, N, S, D, seed=seed)
    assert len(A) == L and len(q) == L + 1
    assert q[0].tolist() == [[0, 0]] and q[L].tolist() == [[N, S]]
    for i, T in enumerate(A):
        Dl, d, Dr = T.shape
        assert d == 4 and Dl == len(q[i]) and Dr == len(q[i + 1]) and max(Dl, Dr) <= D
        allowed = (q[i][:, None, None, :] + SITE_Q[None, :, None, :]
                   == q[i + 1][None, None, :, :]).all(-1)
        assert not np.any(T[~allowed])                  # charge conservation
        # every basis vector of every bond is reached from both sides
        assert (np.abs(T).sum(axis=(1, 2)) > 0).all() and (np.abs(T).sum(axis=(0, 1)) > 0).all()
    B, qb = synth.random_mps(L, N, S, D, seed=seed)
    assert all(np.array_equal(x, y) for x, y in zip(A, B))   # seeded


def test_integrals_symmetries_and_seed():
    I = synth.make_integrals(7, seed=5)
    assert np.allclose(I.h, I.h.T)
    e = I.eri
    for perm in ((1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1)):
        assert np.allclose(e, e.transpose(perm))         # 8-fold chemist symmetry
    # (ij),(kl) supermatrix is positive semidefinite (Cholesky form)
    assert np.linalg.eigvalsh(e.reshape(49, 49)).min() > -1e-12
    J = synth.make_integrals(7, seed=5)
    assert np.array_equal(I.h, J.h) and np.array_equal(I.eri, J.eri)
    K = synth.make_integrals(8, seed=0, n_chol=64, localised_block=True)
    assert np.allclose(np.diag(K.h)[:2], -3.0) and (np.diag(K.h)[2:] > -2.0).all()
