"""Host-side parts of the autograd layer (no GPU): the map from the library's
bond-vector order (vectors grouped by sector, stable within a sector) back
to the caller's order."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
from paper_1902_08489_gb300.grad import _vector_order  # noqa: E402


def test_vector_order_is_the_stable_sector_grouping():
    rng = np.random.default_rng(0)
    sectors = np.array([[0, 0], [1, 1], [1, -1], [2, 0]])
    labels_in = sectors[rng.integers(4, size=40)]
    # the library's order: sectors ascending, the caller's order kept inside each
    order = sorted(range(len(labels_in)), key=lambda x: (tuple(labels_in[x]), x))
    labels_out = labels_in[order]
    p = _vector_order(labels_in, labels_out)
    # out-vector p[x] is in-vector x: same label, and a permutation
    assert np.array_equal(labels_out[p], labels_in)
    assert sorted(p.tolist()) == list(range(len(labels_in)))
    # the k-th vector of a sector maps to the k-th vector of that sector
    assert np.array_equal(np.asarray(order)[p], np.arange(len(labels_in)))


def test_vector_order_round_trip_of_a_site_tensor():
    rng = np.random.default_rng(1)
    ql = np.array([[1, 1], [0, 0], [1, 1]])
    qr = np.array([[2, 0], [1, 1], [2, 0], [1, -1]])
    A = rng.standard_normal((3, 4, 4)) + 1j * rng.standard_normal((3, 4, 4))
    ol = sorted(range(3), key=lambda x: (tuple(ql[x]), x))
    orr = sorted(range(4), key=lambda x: (tuple(qr[x]), x))
    B = A[np.ix_(ol, np.arange(4), orr)]          # the tensor in library order
    pl, pr = _vector_order(ql, ql[ol]), _vector_order(qr, qr[orr])
    assert np.array_equal(B[np.ix_(pl, np.arange(4), pr)], A)
