"""Fiedler orbital ordering: the oracle against closed forms of path graphs,
and the library's host routine (no GPU) against the oracle."""
import numpy as np
import pytest

import synth
from oracle import ordering


def _chain_integrals(L, order, seed):
    """h and eri whose coupling graph is a path through the orbitals in
    `order` (nearest-neighbour hopping and exchange only)."""
    rng = np.random.default_rng(seed)
    h = np.diag(rng.uniform(-2, -0.5, L))
    eri = np.zeros((L, L, L, L))
    for a, b in zip(order[:-1], order[1:]):
        t = rng.uniform(0.5, 1.0)
        h[a, b] = h[b, a] = -t
        k = rng.uniform(0.05, 0.1)
        eri[a, b, b, a] = eri[b, a, a, b] = k
    return h, eri


def test_path_graph_laplacian_closed_form():
    # path graph P_L: lambda_2 = 2 - 2 cos(pi / L), Fiedler vector ~ cos(pi (k + 1/2) / L)
    L = 9
    W = np.zeros((L, L))
    for k in range(L - 1):
        W[k, k + 1] = W[k + 1, k] = 1.0
    lam, V = np.linalg.eigh(ordering.laplacian(W))
    assert abs(lam[1] - (2 - 2 * np.cos(np.pi / L))) < 1e-12
    ref = np.cos(np.pi * (np.arange(L) + 0.5) / L)
    f = V[:, 1]
    assert abs(abs(np.dot(f, ref)) - np.linalg.norm(ref)) < 1e-12


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_oracle_recovers_a_hidden_chain(seed):
    L = 10
    order = np.random.default_rng(100 + seed).permutation(L)
    h, eri = _chain_integrals(L, order, seed)
    perm = ordering.fiedler_order(h, eri)
    assert list(perm) == list(order) or list(perm) == list(order[::-1])


def test_chain_in_exchange_integrals_only_and_forward_sign():
    """Reading of the graph weights: hopping plus exchange (ij|ji).  The
    chain lives only in the exchange integrals, and every Coulomb (ii|jj) is
    the same, so a Coulomb-weighted graph would carry no order.  A chain given
    in input order comes back unreversed: the sign of the Fiedler vector makes
    its correlation with the input order positive."""
    L = 8
    rng = np.random.default_rng(7)
    order = rng.permutation(L)
    for chain, forward in ((order, False), (np.arange(L), True)):
        h = np.diag(rng.uniform(-2, -0.5, L))
        eri = np.zeros((L, L, L, L))
        for i in range(L):
            for j in range(L):
                eri[i, i, j, j] = 0.4
        for a, b in zip(chain[:-1], chain[1:]):
            k = rng.uniform(0.05, 0.1)
            eri[a, b, b, a] = eri[b, a, a, b] = k
        perm = list(ordering.fiedler_order(h, eri))
        if forward:
            assert perm == list(range(L))
        else:
            assert perm == list(chain) or perm == list(chain[::-1])


def test_library_matches_oracle_on_host():
    import paper_1902_08489_gb300 as td
    try:
        td.lib()
    except td.TdmpsError:
        pytest.skip("library not built")
    for L, seed in [(8, 0), (12, 3), (16, 5)]:
        I = synth.make_integrals(L, seed=seed)
        assert list(td.fiedler_order(I.h, I.eri)) == list(ordering.fiedler_order(I.h, I.eri))
    order = np.random.default_rng(7).permutation(11)
    h, eri = _chain_integrals(11, order, 7)
    assert list(td.fiedler_order(h, eri)) == list(ordering.fiedler_order(h, eri))
    # the permuted integrals are those of the reordered orbitals
    p = td.fiedler_order(h, eri)
    h2, e2 = td.permute_integrals(h, eri, p)
    assert h2[0, 1] == h[p[0], p[1]] and e2[0, 1, 1, 0] == eri[p[0], p[1], p[1], p[0]]


def test_library_rejects_bad_input_on_host():
    import paper_1902_08489_gb300 as td
    try:
        td.lib()
    except td.TdmpsError:
        pytest.skip("library not built")
    I = synth.make_integrals(5, seed=9)
    h = I.h.copy()
    h[1, 2] = np.nan
    with pytest.raises(td.TdmpsError) as e:
        td.fiedler_order(h, I.eri)
    assert e.value.name == "NONFINITE"
    # L = 65 is rejected before the integral arrays are read
    with pytest.raises(td.TdmpsError) as e:
        td.fiedler_order(np.zeros((65, 65)), np.zeros(1))
    assert e.value.name == "INVALID_ARG"
    # one and two orbitals have a single ordering
    assert list(td.fiedler_order(I.h[:2, :2], I.eri[:2, :2, :2, :2])) == [0, 1]


def test_weights_by_hand():
    # w_ij = (|h_ij| + |h_ji| + |K_ij| + |K_ji|) / 2 with the exchange integral
    # K_ij = (ij|ji), zero diagonal; the Coulomb integrals (ii|jj) do not enter
    from oracle import ordering as oo
    h = np.array([[-1.0, 0.3, 0.0], [0.3, -0.5, -0.2], [0.0, -0.2, 0.1]])
    eri = np.zeros((3, 3, 3, 3))
    eri[0, 1, 1, 0] = eri[1, 0, 0, 1] = 0.05
    eri[0, 2, 2, 0] = 0.02
    eri[2, 0, 0, 2] = -0.04
    eri[1, 1, 2, 2] = eri[2, 2, 1, 1] = 0.7     # Coulomb: ignored
    expect = np.array([[0.0, 0.35, 0.03], [0.35, 0.0, 0.2], [0.03, 0.2, 0.0]])
    assert np.allclose(oo.weights(h, eri), expect, atol=1e-15, rtol=0)
